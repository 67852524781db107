"""B300 electrostatic PIC hot path: Python binding of the C ABI in include/ap_pic.h.

Argument marshalling only: every step of the cycle runs in the CUDA kernels of
libap_pic.so.  If the library is missing or cannot be loaded, importing this
package's calls raises; there is no other execution path.

PyTorch supplies device memory (its caching allocator, through the ABI's
allocator callbacks) and the CUDA stream.
"""

from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libap_pic.so")

AP_PIC_OK = 0
STATUS = {
    0: "AP_PIC_OK", -1: "AP_PIC_ERR_ARG", -2: "AP_PIC_ERR_UNSUPPORTED", -3: "AP_PIC_ERR_NOMEM",
    -4: "AP_PIC_ERR_CUDA", -5: "AP_PIC_ERR_NOT_CONVERGED", -6: "AP_PIC_ERR_BOUNDS",
    -7: "AP_PIC_ERR_STATE", -8: "AP_PIC_ERR_TOO_LARGE",
}
AP_PIC_NOALLOC_MAX_NP = 1 << 20
AP_PIC_BC_PERIODIC = 0
AP_PIC_FP32_CELLOFF = 0
AP_PIC_FP64_PLAIN = 1
AP_PIC_SOLVER_CG = 0
AP_PIC_SOLVER_FFT = 1
AP_PIC_FFT_MAX_N = 4096
AP_PIC_PUSHER_BORIS = 0
AP_PIC_PUSHER_HIGUERA_CARY = 1
AP_PIC_LOAD_NO_HALFPUSH = 1

# Every symbol the header declares (checked by the CPU test of the library's exports).
EXPORTS = [
    "ap_pic_config_default", "ap_pic_create", "ap_pic_get_config", "ap_pic_destroy", "ap_pic_load",
    "ap_pic_load_state", "ap_pic_gather_push", "ap_pic_deposit", "ap_pic_push_deposit",
    "ap_pic_solve_field", "ap_pic_sort", "ap_pic_step", "ap_pic_get_rho", "ap_pic_get_E",
    "ap_pic_get_phi", "ap_pic_get_rho_fx", "ap_pic_get_particles", "ap_pic_get_velocities_f64",
    "ap_pic_get_perm", "ap_pic_get_diag", "ap_pic_set_timing", "ap_pic_get_timing",
    "ap_pic_kernel_launches", "ap_pic_num_particles", "ap_pic_last_error", "ap_pic_version",
    "ap_pic_sort_perm_noalloc", "ap_pic_set_collisions", "ap_pic_collide", "ap_pic_get_B",
    "ap_pic_set_current",
    "ap_pic_batch_default_tuning", "ap_pic_batch_create", "ap_pic_batch_destroy",
    "ap_pic_batch_load", "ap_pic_batch_step", "ap_pic_batch_push_deposit", "ap_pic_batch_sort",
    "ap_pic_batch_solve_field", "ap_pic_batch_set_tuning",
    "ap_pic_batch_get_tuning", "ap_pic_batch_autotune", "ap_pic_batch_get_rho",
    "ap_pic_batch_get_E", "ap_pic_batch_get_particles", "ap_pic_batch_get_perm",
    "ap_pic_batch_get_diag", "ap_pic_batch_num_particles", "ap_pic_batch_last_error",
]
STAGES = ["push_deposit", "rho", "sort", "field", "diag"]
NSTAGES = 8


class ap_pic_config(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
        ("dt", ctypes.c_double), ("q", ctypes.c_double), ("m", ctypes.c_double),
        ("weight", ctypes.c_double), ("rho_background", ctypes.c_double),
        ("E0", ctypes.c_double * 3), ("B0", ctypes.c_double * 3), ("bc", ctypes.c_int),
        ("precision", ctypes.c_int), ("nv", ctypes.c_int), ("sort_every", ctypes.c_int),
        ("fx_bits", ctypes.c_int), ("cg_rtol", ctypes.c_double), ("cg_maxit", ctypes.c_int),
        ("brick", ctypes.c_int * 3), ("diag_every", ctypes.c_int), ("solver", ctypes.c_int),
        ("pusher", ctypes.c_int), ("c_light", ctypes.c_double), ("em", ctypes.c_int),
        ("em_boundary", ctypes.c_int), ("pml_cells", ctypes.c_int),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class ap_pic_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class ap_pic_diag(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("t", ctypes.c_double), ("np", ctypes.c_int64),
        ("fx_bits", ctypes.c_int), ("charge_fx_sum", ctypes.c_int64),
        ("total_charge", ctypes.c_double), ("kinetic", ctypes.c_double),
        ("field_energy", ctypes.c_double), ("momentum", ctypes.c_double * 3),
        ("cg_iters", ctypes.c_int), ("cg_relres", ctypes.c_double), ("error_flags", ctypes.c_int),
        ("mcc_counts", ctypes.c_int64 * 3),
    ]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k in ("momentum", "mcc_counts") else getattr(self, k))
                for k, _ in self._fields_}


class ap_pic_mcc(ctypes.Structure):
    _fields_ = [("density", ctypes.c_double), ("sigma_el", ctypes.c_double),
                ("sigma_exc", ctypes.c_double), ("eps_exc", ctypes.c_double),
                ("mass_ratio", ctypes.c_double), ("vmax", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class ap_pic_batch_tuning(ctypes.Structure):
    _fields_ = [("pass_ctas_per_sm", ctypes.c_int), ("item_cells", ctypes.c_int),
                ("sort_every", ctypes.c_int), ("cg_iters_per_graph", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("pass_threads", ctypes.c_int),
                ("pass_per_thread", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded CUDA library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2608_15249_b300/build.py "
                               "(nvcc, sm_103a) first")
        _lib = ctypes.CDLL(LIB_PATH)
        _declare(_lib)
    return _lib


def _declare(L):
    P, I64, I, U = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint
    cfgp = ctypes.POINTER(ap_pic_config)
    L.ap_pic_config_default.argtypes = [cfgp]
    L.ap_pic_config_default.restype = None
    L.ap_pic_create.argtypes = [cfgp, ctypes.POINTER(ap_pic_allocator), P, ctypes.POINTER(P)]
    L.ap_pic_get_config.argtypes = [P, cfgp]
    L.ap_pic_destroy.argtypes = [P]
    L.ap_pic_load.argtypes = [P, I64, P, P, U]
    L.ap_pic_load_state.argtypes = [P, I64, P, P, P, U]
    for name in ("ap_pic_gather_push", "ap_pic_deposit", "ap_pic_push_deposit",
                 "ap_pic_solve_field", "ap_pic_sort"):
        getattr(L, name).argtypes = [P]
    L.ap_pic_step.argtypes = [P, I]
    for name in ("ap_pic_get_rho", "ap_pic_get_E", "ap_pic_get_phi", "ap_pic_get_rho_fx",
                 "ap_pic_get_velocities_f64", "ap_pic_get_perm"):
        getattr(L, name).argtypes = [P, P]
    L.ap_pic_get_particles.argtypes = [P, P, P, P, P]
    L.ap_pic_get_diag.argtypes = [P, ctypes.POINTER(ap_pic_diag)]
    L.ap_pic_set_timing.argtypes = [P, I]
    L.ap_pic_set_collisions.argtypes = [P, ctypes.POINTER(ap_pic_mcc)]
    L.ap_pic_collide.argtypes = [P]
    L.ap_pic_get_B.argtypes = [P, P]
    L.ap_pic_set_current.argtypes = [P, P]
    L.ap_pic_get_timing.argtypes = [P, P, P]
    L.ap_pic_kernel_launches.argtypes = []
    L.ap_pic_kernel_launches.restype = I64
    L.ap_pic_num_particles.argtypes = [P]
    L.ap_pic_num_particles.restype = I64
    L.ap_pic_last_error.argtypes = [P]
    L.ap_pic_last_error.restype = ctypes.c_char_p
    L.ap_pic_sort_perm_noalloc.argtypes = [I, P, P, I64, P, P, P]
    tunp = ctypes.POINTER(ap_pic_batch_tuning)
    L.ap_pic_batch_default_tuning.argtypes = [tunp]
    L.ap_pic_batch_default_tuning.restype = None
    L.ap_pic_batch_create.argtypes = [I, P, ctypes.POINTER(ap_pic_allocator), P, ctypes.POINTER(P)]
    L.ap_pic_batch_destroy.argtypes = [P]
    L.ap_pic_batch_load.argtypes = [P, P, P, P, U]
    L.ap_pic_batch_step.argtypes = [P, I]
    for name in ("ap_pic_batch_push_deposit", "ap_pic_batch_sort", "ap_pic_batch_solve_field"):
        getattr(L, name).argtypes = [P]
        getattr(L, name).restype = I
    L.ap_pic_batch_set_tuning.argtypes = [P, tunp]
    L.ap_pic_batch_get_tuning.argtypes = [P, tunp]
    L.ap_pic_batch_autotune.argtypes = [P, I, ctypes.c_char_p]
    for name in ("ap_pic_batch_get_rho", "ap_pic_batch_get_E", "ap_pic_batch_get_perm"):
        getattr(L, name).argtypes = [P, I, P]
    L.ap_pic_batch_get_particles.argtypes = [P, I, P, P, P, P]
    L.ap_pic_batch_get_diag.argtypes = [P, I, ctypes.POINTER(ap_pic_diag)]
    L.ap_pic_batch_num_particles.argtypes = [P, I]
    L.ap_pic_batch_num_particles.restype = I64
    L.ap_pic_batch_last_error.argtypes = [P]
    L.ap_pic_batch_last_error.restype = ctypes.c_char_p
    L.ap_pic_version.argtypes = []
    L.ap_pic_version.restype = ctypes.c_char_p


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def make_config(ndim, n, dx=(1.0, 1.0, 1.0), dt=0.1, q=-1.0, m=1.0, weight=1.0,
                rho_background=None, E0=(0, 0, 0), B0=(0, 0, 0), nv=None,
                precision=AP_PIC_FP32_CELLOFF, sort_every=20, fx_bits=0, cg_rtol=0.0,
                cg_maxit=0, brick=(0, 0, 0), diag_every=0,
                solver=AP_PIC_SOLVER_CG, pusher=AP_PIC_PUSHER_BORIS,
                c_light=0.0, em=0, em_boundary=0, pml_cells=0) -> ap_pic_config:
    c = ap_pic_config()
    lib().ap_pic_config_default(ctypes.byref(c))
    c.ndim = ndim
    nn = list(n) + [1] * 3
    dd = list(dx) + [1.0] * 3
    for a in range(3):
        c.n[a] = int(nn[a]) if a < ndim else 1
        c.dx[a] = float(dd[a]) if a < ndim else 1.0
        c.E0[a] = float((list(E0) + [0, 0, 0])[a])
        c.B0[a] = float((list(B0) + [0, 0, 0])[a])
        c.brick[a] = int((list(brick) + [0, 0, 0])[a])
    c.dt, c.q, c.m, c.weight = float(dt), float(q), float(m), float(weight)
    c.rho_background = math.nan if rho_background is None else float(rho_background)
    c.nv = int(nv if nv is not None else ndim)
    c.precision = int(precision)
    c.sort_every = int(sort_every)
    c.fx_bits = int(fx_bits)
    c.cg_rtol = float(cg_rtol)
    c.cg_maxit = int(cg_maxit)
    c.diag_every = int(diag_every)
    c.solver = int(solver)
    c.pusher = int(pusher)
    c.c_light = float(c_light)
    c.em = int(em)
    c.em_boundary = int(em_boundary)
    c.pml_cells = int(pml_cells)
    return c


class _TorchAllocator:
    """ABI allocator callbacks backed by PyTorch's CUDA caching allocator."""

    def __init__(self):
        import torch

        self._torch = torch
        self._dev = torch.cuda.current_device()
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = ap_pic_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), self._dev)
        except Exception:  # noqa: BLE001  (reported to the library as NULL -> AP_PIC_ERR_NOMEM)
            return None

    def _do_free(self, ptr, nbytes, ctx):
        self._torch.cuda.caching_allocator_delete(ptr)


class Pic:
    """One PIC instance: a handle of the C library plus numpy marshalling."""

    def __init__(self, cfg: ap_pic_config, stream=None, use_torch_allocator=True):
        self._lib = lib()
        self.cfg = cfg
        self.ndim, self.nv = cfg.ndim, cfg.nv
        self.cells = int(np.prod([cfg.n[a] for a in range(cfg.ndim)]))
        self._alloc = None
        allocp = None
        if use_torch_allocator:
            self._alloc = _TorchAllocator()
            allocp = ctypes.byref(self._alloc.struct)
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream().cuda_stream
            except Exception:  # noqa: BLE001
                stream = 0
        self.stream = stream
        h = ctypes.c_void_p()
        st = self._lib.ap_pic_create(ctypes.byref(cfg), allocp, ctypes.c_void_p(stream or 0),
                                     ctypes.byref(h))
        self.h = h
        if st != AP_PIC_OK:
            msg = self.last_error()
            self._lib.ap_pic_destroy(h)
            self.h = None
            raise PicError(st, msg)
        resolved = ap_pic_config()
        self._check(self._lib.ap_pic_get_config(self.h, ctypes.byref(resolved)))
        self.cfg = resolved

    # -- plumbing
    def last_error(self):
        return self._lib.ap_pic_last_error(self.h).decode() if self.h else ""

    def _check(self, st):
        if st != AP_PIC_OK:
            raise PicError(st, self.last_error())

    def close(self):
        if getattr(self, "h", None):
            self._lib.ap_pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls (names follow the C ABI)
    @property
    def np(self):
        return int(self._lib.ap_pic_num_particles(self.h))

    def load(self, x, v, half_push=True):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        assert x.shape[1] == self.ndim and v.shape[1] == self.nv and x.shape[0] == v.shape[0]
        flags = 0 if half_push else AP_PIC_LOAD_NO_HALFPUSH
        self._check(self._lib.ap_pic_load(self.h, x.shape[0], _ptr(x), _ptr(v), flags))
        return self

    def load_ptr(self, npart, x_ptr, v_ptr, half_push=True):
        """Load from raw host pointers (e.g. pinned buffers)."""
        flags = 0 if half_push else AP_PIC_LOAD_NO_HALFPUSH
        self._check(self._lib.ap_pic_load(self.h, int(npart), ctypes.c_void_p(x_ptr),
                                          ctypes.c_void_p(v_ptr), flags))
        return self

    def load_state(self, cell, off, v, half_push=False):
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        off = np.ascontiguousarray(off, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        flags = 0 if half_push else AP_PIC_LOAD_NO_HALFPUSH
        self._check(self._lib.ap_pic_load_state(self.h, cell.size, _ptr(cell), _ptr(off), _ptr(v),
                                                flags))
        return self

    def gather_push(self):
        self._check(self._lib.ap_pic_gather_push(self.h))

    def deposit(self):
        self._check(self._lib.ap_pic_deposit(self.h))

    def push_deposit(self):
        self._check(self._lib.ap_pic_push_deposit(self.h))

    def solve_field(self):
        self._check(self._lib.ap_pic_solve_field(self.h))

    def set_collisions(self, density=None, sigma_el=0.0, sigma_exc=0.0, eps_exc=0.0,
                       mass_ratio=0.0, vmax=1.0, seed=0):
        """Null-collision Monte Carlo (before load); density=None disables it."""
        if density is None:
            self._check(self._lib.ap_pic_set_collisions(self.h, None))
            return self
        c = ap_pic_mcc(float(density), float(sigma_el), float(sigma_exc), float(eps_exc),
                       float(mass_ratio), float(vmax), int(seed))
        self._check(self._lib.ap_pic_set_collisions(self.h, ctypes.byref(c)))
        return self

    def collide(self):
        self._check(self._lib.ap_pic_collide(self.h))

    def sort(self):
        self._check(self._lib.ap_pic_sort(self.h))

    def step(self, nsteps=1):
        self._check(self._lib.ap_pic_step(self.h, int(nsteps)))

    def get_rho(self):
        out = np.empty(self.cells, np.float64)
        self._check(self._lib.ap_pic_get_rho(self.h, _ptr(out)))
        return out

    def get_rho_fx(self):
        out = np.empty(self.cells, np.int64)
        self._check(self._lib.ap_pic_get_rho_fx(self.h, _ptr(out)))
        return out

    def get_E(self):
        """ndim x cells (node-centred), or 3 x cells Yee-staggered with em = 1."""
        comps = 3 if self.cfg.em else self.ndim
        out = np.empty(comps * self.cells, np.float64)
        self._check(self._lib.ap_pic_get_E(self.h, _ptr(out)))
        return out

    def set_current(self, J):
        """Prescribed current (3 x cells, staggered like E) for the following
        electromagnetic steps; None clears it."""
        if J is None:
            self._check(self._lib.ap_pic_set_current(self.h, None))
            return
        J = np.ascontiguousarray(J, dtype=np.float64)
        assert J.size == 3 * self.cells
        self._check(self._lib.ap_pic_set_current(self.h, _ptr(J)))

    def get_B(self):
        """3 x cells Yee-staggered magnetic field (em = 1)."""
        out = np.empty(3 * self.cells, np.float64)
        self._check(self._lib.ap_pic_get_B(self.h, _ptr(out)))
        return out

    def get_phi(self):
        out = np.empty(self.cells, np.float64)
        self._check(self._lib.ap_pic_get_phi(self.h, _ptr(out)))
        return out

    def get_particles(self, positions=True):
        n = self.np
        cell = np.empty(n, np.int32)
        off = np.empty((n, self.ndim), np.float32)
        v = np.empty((n, self.nv), np.float32)
        x = np.empty((n, self.ndim), np.float64) if positions else None
        self._check(self._lib.ap_pic_get_particles(self.h, _ptr(cell), _ptr(off), _ptr(v),
                                                   _ptr(x)))
        return cell, off, v, x

    def get_velocities_f64(self):
        out = np.empty((self.np, self.nv), np.float64)
        self._check(self._lib.ap_pic_get_velocities_f64(self.h, _ptr(out)))
        return out

    def get_perm(self):
        out = np.empty(self.np, np.int64)
        self._check(self._lib.ap_pic_get_perm(self.h, _ptr(out)))
        return out

    def set_timing(self, enable=True):
        self._check(self._lib.ap_pic_set_timing(self.h, 1 if enable else 0))

    def get_timing(self) -> dict:
        """Per stage: (total ms, occurrences) since set_timing(True)."""
        ms = np.zeros(NSTAGES, np.float64)
        n = np.zeros(NSTAGES, np.int64)
        self._check(self._lib.ap_pic_get_timing(self.h, _ptr(ms), _ptr(n)))
        return {name: (float(ms[k]), int(n[k])) for k, name in enumerate(STAGES)}

    def get_config(self) -> ap_pic_config:
        c = ap_pic_config()
        self._check(self._lib.ap_pic_get_config(self.h, ctypes.byref(c)))
        return c

    def get_diag(self) -> dict:
        d = ap_pic_diag()
        self._check(self._lib.ap_pic_get_diag(self.h, ctypes.byref(d)))
        return d.as_dict()


def from_workload(w, stream=None, **over) -> Pic:
    """A Pic configured for a `workloads.Workload` (positions not loaded yet)."""
    kw = dict(ndim=w.ndim, n=w.n, dx=w.dx, dt=w.dt, q=w.q, m=w.m, weight=w.weight, B0=w.B0,
              E0=w.E0, nv=w.nv, sort_every=w.sort_every)
    kw.update(over)
    return Pic(make_config(**kw), stream=stream)


class Batch:
    """Many independent instances advanced together (the C ABI's ap_pic_batch_*)."""

    def __init__(self, cfgs, stream=None, use_torch_allocator=True):
        self._lib = lib()
        self.cfgs = list(cfgs)
        self.count = len(self.cfgs)
        arr = (ap_pic_config * self.count)(*self.cfgs)
        self._alloc = _TorchAllocator() if use_torch_allocator else None
        allocp = ctypes.byref(self._alloc.struct) if self._alloc else None
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream().cuda_stream
            except Exception:  # noqa: BLE001
                stream = 0
        h = ctypes.c_void_p()
        st = self._lib.ap_pic_batch_create(self.count, arr, allocp, ctypes.c_void_p(stream or 0),
                                           ctypes.byref(h))
        self.h = h
        if st != AP_PIC_OK:
            msg = self.last_error()
            self._lib.ap_pic_batch_destroy(h)
            self.h = None
            raise PicError(st, msg)

    def last_error(self):
        return self._lib.ap_pic_batch_last_error(self.h).decode() if self.h else ""

    def _check(self, st):
        if st != AP_PIC_OK:
            raise PicError(st, self.last_error())

    def close(self):
        if getattr(self, "h", None):
            self._lib.ap_pic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def load(self, xs, vs, half_push=True):
        xs = [np.ascontiguousarray(x, dtype=np.float64) for x in xs]
        vs = [np.ascontiguousarray(v, dtype=np.float64) for v in vs]
        nps = (ctypes.c_int64 * self.count)(*[x.shape[0] for x in xs])
        xp = (ctypes.c_void_p * self.count)(*[x.ctypes.data for x in xs])
        vp = (ctypes.c_void_p * self.count)(*[v.ctypes.data for v in vs])
        self._keep = (xs, vs)
        flags = 0 if half_push else AP_PIC_LOAD_NO_HALFPUSH
        self._check(self._lib.ap_pic_batch_load(self.h, nps, xp, vp, flags))
        self._keep = None
        return self

    def step(self, nsteps=1):
        self._check(self._lib.ap_pic_batch_step(self.h, int(nsteps)))

    def push_deposit(self):
        self._check(self._lib.ap_pic_batch_push_deposit(self.h))

    def sort(self):
        self._check(self._lib.ap_pic_batch_sort(self.h))

    def solve_field(self):
        self._check(self._lib.ap_pic_batch_solve_field(self.h))

    def get_tuning(self):
        t = ap_pic_batch_tuning()
        self._check(self._lib.ap_pic_batch_get_tuning(self.h, ctypes.byref(t)))
        return t

    def set_tuning(self, **kw):
        t = self.get_tuning()
        for k, v in kw.items():
            setattr(t, k, int(v))
        self._check(self._lib.ap_pic_batch_set_tuning(self.h, ctypes.byref(t)))

    def autotune(self, steps_per_trial=4, cache_path=None):
        cp = cache_path.encode() if cache_path else None
        self._check(self._lib.ap_pic_batch_autotune(self.h, int(steps_per_trial), cp))
        return self.get_tuning().as_dict()

    def num_particles(self, i):
        return int(self._lib.ap_pic_batch_num_particles(self.h, i))

    def _cells(self, i):
        c = self.cfgs[i]
        return int(np.prod([c.n[a] for a in range(c.ndim)]))

    def get_rho(self, i):
        out = np.empty(self._cells(i), np.float64)
        self._check(self._lib.ap_pic_batch_get_rho(self.h, i, _ptr(out)))
        return out

    def get_E(self, i):
        out = np.empty(self.cfgs[i].ndim * self._cells(i), np.float64)
        self._check(self._lib.ap_pic_batch_get_E(self.h, i, _ptr(out)))
        return out

    def get_particles(self, i):
        n, nd = self.num_particles(i), self.cfgs[i].ndim
        cell = np.empty(n, np.int32)
        off = np.empty((n, nd), np.float32)
        v = np.empty((n, 2), np.float32)
        x = np.empty((n, nd), np.float64)
        self._check(self._lib.ap_pic_batch_get_particles(self.h, i, _ptr(cell), _ptr(off),
                                                         _ptr(v), _ptr(x)))
        return cell, off, v, x

    def get_perm(self, i):
        out = np.empty(self.num_particles(i), np.int64)
        self._check(self._lib.ap_pic_batch_get_perm(self.h, i, _ptr(out)))
        return out

    def get_diag(self, i):
        d = ap_pic_diag()
        self._check(self._lib.ap_pic_batch_get_diag(self.h, i, ctypes.byref(d)))
        return d.as_dict()


def batch_from_workloads(ws, stream=None, **over):
    """A Batch configured for a list of `workloads.Workload` (not loaded yet)."""
    cfgs = []
    for w in ws:
        kw = dict(ndim=w.ndim, n=w.n, dx=w.dx, dt=w.dt, q=w.q, m=w.m, weight=w.weight,
                  E0=w.E0, nv=w.nv, sort_every=w.sort_every)
        kw.update(over)
        cfgs.append(make_config(**kw))
    return Batch(cfgs, stream=stream)


def kernel_launches() -> int:
    return int(lib().ap_pic_kernel_launches())


def version() -> str:
    return lib().ap_pic_version().decode()
