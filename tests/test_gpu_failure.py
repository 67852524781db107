"""Failure and restart paths of the C ABI on host-safe inputs: no kernel is made to
fault, trap or hang.

* a field solve capped at cg_maxit = 1 returns AP_PIC_ERR_NOT_CONVERGED and latches
  the solve's flag in the diagnostics;
* non-finite loaded positions or velocities return AP_PIC_ERR_BOUNDS, leave the handle
  unloaded, and stay reported (errors are sticky until ap_pic_destroy);
* an allocator callback that returns NULL gives AP_PIC_ERR_NOMEM at whichever
  allocation it refuses, and ap_pic_destroy then returns every block it was given;
* a checkpoint (ap_pic_get_particles) restored with ap_pic_load_state continues
  exactly as the uninterrupted run: bit for bit with the spectral solve, within the
  solve's tolerance with the CG (which warm-starts from the previous potential).
"""

import ctypes
import math

import numpy as np
import pytest

from workloads import plasma

pytestmark = pytest.mark.gpu

EF_CG = 2


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2608_15249_b300 as pk
    pk.lib()
    return pk, torch


def _w():
    return plasma.maxwellian_box(2, (32, 24), ppc=16, nv=2, dt=0.1, seed=101)


def test_cg_cap_reports_not_converged(env):
    pk, _ = env
    w = _w()
    g = pk.from_workload(w, cg_maxit=1, cg_rtol=1e-7)
    with pytest.raises(pk.PicError) as ei:
        g.load(w.x, w.v)
    assert ei.value.status == -5            # AP_PIC_ERR_NOT_CONVERGED
    d = g.get_diag()
    assert d["error_flags"] & EF_CG
    assert d["cg_iters"] <= 2
    g.close()


@pytest.mark.parametrize("where,value", [("x", math.nan), ("x", math.inf), ("v", math.nan),
                                         ("v", -math.inf)])
def test_non_finite_load_is_rejected(env, where, value):
    pk, _ = env
    w = _w()
    x, v = w.x.copy(), w.v.copy()
    (x if where == "x" else v)[17, 1] = value
    g = pk.from_workload(w)
    with pytest.raises(pk.PicError) as ei:
        g.load(x, v)
    assert ei.value.status == -6            # AP_PIC_ERR_BOUNDS
    with pytest.raises(pk.PicError) as ei:
        g.step(1)                           # nothing was loaded
    assert ei.value.status == -7            # AP_PIC_ERR_STATE
    with pytest.raises(pk.PicError) as ei:
        g.load(w.x, w.v)                    # sticky until destroy
    assert ei.value.status == -6
    g.close()
    h = pk.from_workload(w).load(w.x, w.v)  # a new handle is unaffected
    h.step(2)
    h.close()


class _CountingAllocator:
    """ABI allocator callbacks over PyTorch's caching allocator that refuse (return
    NULL) once `budget` blocks have been handed out, and track the live blocks."""

    def __init__(self, pk, torch, budget):
        self.torch, self.budget, self.given = torch, budget, 0
        self.live = {}
        self.dev = torch.cuda.current_device()
        self._a = pk.ALLOC_FN(self._alloc)
        self._f = pk.FREE_FN(self._free)
        self.struct = pk.ap_pic_allocator(self._a, self._f, None)

    def _alloc(self, nbytes, ctx):
        if self.budget is not None and self.given >= self.budget:
            return None
        self.given += 1
        ptr = self.torch.cuda.caching_allocator_alloc(int(nbytes), self.dev)
        self.live[ptr] = int(nbytes)
        return ptr

    def _free(self, ptr, nbytes, ctx):
        assert ptr in self.live and self.live[ptr] == nbytes
        del self.live[ptr]
        self.torch.cuda.caching_allocator_delete(ptr)


def _create_and_load(pk, torch, w, budget):
    L = pk.lib()
    al = _CountingAllocator(pk, torch, budget)
    cfg = pk.make_config(ndim=w.ndim, n=w.n, dx=w.dx, dt=w.dt, weight=w.weight, nv=w.nv,
                         solver=pk.AP_PIC_SOLVER_FFT)
    h = ctypes.c_void_p()
    st = L.ap_pic_create(ctypes.byref(cfg), ctypes.byref(al.struct),
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                         ctypes.byref(h))
    if st == 0:
        x = np.ascontiguousarray(w.x)
        v = np.ascontiguousarray(w.v)
        st = L.ap_pic_load(h, w.np_, ctypes.c_void_p(x.ctypes.data),
                           ctypes.c_void_p(v.ctypes.data), 0)
        if st == 0:
            st = L.ap_pic_step(h, 2)
    L.ap_pic_destroy(h)
    torch.cuda.synchronize()
    return st, al


def test_refused_allocation_gives_nomem_and_leaks_nothing(env):
    pk, torch = env
    w = _w()
    st, al = _create_and_load(pk, torch, w, None)
    assert st == 0 and not al.live
    total = al.given
    assert total >= 3
    for budget in sorted(set([0, 1, total // 2, total - 1])):
        st, al = _create_and_load(pk, torch, w, budget)
        assert st == -3, (budget, st)         # AP_PIC_ERR_NOMEM
        assert not al.live, (budget, al.live)  # everything handed out was returned


@pytest.mark.parametrize("solver", ["fft", "cg"])
def test_checkpoint_restart_continues_the_run(env, solver):
    """Run A: load, 6 steps (sorted at steps 3 and 6), read the state, 5 more steps.
    Run B: load_state(A's state after 6 steps, no half push), 5 steps.  The sort
    cadence lines up because the checkpoint falls on a sort (B's restore sorts an
    already sorted array: the identity)."""
    pk, _ = env
    w = plasma.two_stream_2d(n=(64, 48), ppc=16, mode=(2, 1), seed=102)
    sv = pk.AP_PIC_SOLVER_FFT if solver == "fft" else pk.AP_PIC_SOLVER_CG
    a = pk.from_workload(w, sort_every=3, solver=sv, cg_rtol=1e-7).load(w.x, w.v)
    a.step(6)
    cell, off, v, _ = a.get_particles(positions=False)
    b = pk.from_workload(w, sort_every=3, solver=sv, cg_rtol=1e-7)
    b.load_state(cell, off, v, half_push=False)
    np.testing.assert_array_equal(b.get_perm(), np.arange(w.np_))
    a.step(5)
    b.step(5)
    ta, tb = a.get_particles(), b.get_particles()
    if solver == "fft":
        for xa, xb in zip(ta, tb):
            np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(a.get_rho_fx(), b.get_rho_fx())
        np.testing.assert_array_equal(a.get_E(), b.get_E())
        da, db = a.get_diag(), b.get_diag()
        assert da["kinetic"] == db["kinetic"] and da["momentum"] == db["momentum"]
    else:
        L = np.asarray(w.L[:2])
        dist = np.abs(ta[3] - tb[3])
        assert np.minimum(dist, L - dist).max() <= 1e-5   # positions, in cells (dx = 1)
        assert np.abs(ta[2] - tb[2]).max() <= 1e-5 * np.abs(ta[2]).max()
        Ea = a.get_E()
        assert np.abs(Ea - b.get_E()).max() <= 1e-5 * np.abs(Ea).max()
    a.close()
    b.close()
