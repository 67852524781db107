"""The no-allocation sort entry point (GPU).

ap_pic_sort_perm_noalloc serves callers that may not call cudaMalloc (a host
framework that owns the device's memory through its own pool, or a hot loop that
cannot afford cudaMalloc/cudaFree's device-wide synchronisation).  Its scratch is a
fixed array in device global memory shared by every call.  It must give exactly
the permutation of the allocating entry point, ap_pic_sort, on the same cells --
on two calls in a row, so that the second call also proves that whatever the
first left in the shared scratch does not leak into its result.

This file sorts last (pytest collects it after the other test files), so a run
that stops at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

from workloads import plasma

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2608_15249_b300 as pk
    pk.lib()
    return pk, torch


def _call(pk, ndim, n, brick, npart, cell_ptr, perm_ptr, stream):
    n3 = (ctypes.c_int * 3)(*(list(n) + [1, 1, 1])[:3])
    b3 = (ctypes.c_int * 3)(*(list(brick) + [1, 1, 1])[:3])
    return pk.lib().ap_pic_sort_perm_noalloc(ndim, n3, b3, int(npart), ctypes.c_void_p(cell_ptr),
                                             ctypes.c_void_p(perm_ptr), ctypes.c_void_p(stream))


def test_noalloc_sort_matches_allocating_sort(env):
    pk, torch = env
    stream = torch.cuda.current_stream()
    # two calls in a row, of different sizes and grids, each checked exactly
    cases = [plasma.maxwellian_box(2, (40, 36), ppc=24, nv=2, seed=51),
             plasma.maxwellian_box(3, (12, 10, 9), ppc=9, nv=3, seed=52)]
    for w in cases:
        g = pk.from_workload(w, sort_every=0).load(w.x, w.v)
        g.step(3)  # move the particles away from the order the load left them in
        cell, _, _, _ = g.get_particles(positions=False)
        g.sort()
        want = g.get_perm()
        brick = [g.cfg.brick[a] for a in range(3)]
        d_cell = torch.from_numpy(cell).to("cuda")
        d_perm = torch.full((w.np_,), -1, dtype=torch.int32, device="cuda")
        st = _call(pk, w.ndim, w.n, brick, w.np_, d_cell.data_ptr(), d_perm.data_ptr(),
                   stream.cuda_stream)
        assert st == pk.AP_PIC_OK, st
        torch.cuda.synchronize()
        np.testing.assert_array_equal(d_perm.cpu().numpy().astype(np.int64), want)
        g.close()


def _noalloc_vs_sort(pk, torch, w, brick_arg, stream_ptr, steps=3):
    g = pk.from_workload(w, sort_every=0).load(w.x, w.v)
    g.step(steps)
    cell, _, _, _ = g.get_particles(positions=False)
    g.sort()
    want = g.get_perm()
    g.close()
    d_cell = torch.from_numpy(cell).to("cuda")
    d_perm = torch.full((w.np_,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    st = _call(pk, w.ndim, w.n, brick_arg, w.np_, d_cell.data_ptr(), d_perm.data_ptr(),
               stream_ptr)
    assert st == pk.AP_PIC_OK, st
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d_perm.cpu().numpy().astype(np.int64), want)


@pytest.mark.parametrize("case", ["1d_default_brick", "2d_default_brick_stream0",
                                  "2d_capacity_10bit_digits"])
def test_noalloc_defaults_capacity_and_default_stream(env, case):
    """brick (0, 0, 0) takes the library default (ap_pic_sort's, on a handle created
    with its default brick); a 1D grid; a call on the legacy default stream (NULL);
    and exactly AP_PIC_NOALLOC_MAX_NP particles on a 1024 x 1024 grid, whose 20-bit
    keys sort in two 10-bit digit passes, so the per-tile histograms fill the fixed
    array to its end."""
    pk, torch = env
    stream = torch.cuda.current_stream().cuda_stream
    if case == "1d_default_brick":
        w = plasma.maxwellian_box(1, (1000,), ppc=40, nv=1, seed=53)
        _noalloc_vs_sort(pk, torch, w, (0, 0, 0), stream)
    elif case == "2d_default_brick_stream0":
        w = plasma.maxwellian_box(2, (70, 50), ppc=12, nv=2, seed=54)
        _noalloc_vs_sort(pk, torch, w, (0, 0, 0), 0)
    else:
        w = plasma.maxwellian_box(2, (1024, 1024), ppc=1, nv=2, seed=55)
        assert w.np_ == pk.AP_PIC_NOALLOC_MAX_NP
        _noalloc_vs_sort(pk, torch, w, (0, 0, 0), stream, steps=2)


def test_noalloc_rejects_more_than_its_capacity(env):
    pk, torch = env
    st = _call(pk, 2, (8, 8), (0, 0), pk.AP_PIC_NOALLOC_MAX_NP + 1, 0, 0, 0)
    assert st == -8  # AP_PIC_ERR_TOO_LARGE, before any device work
