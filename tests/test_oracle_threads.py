"""The oracle's optional threading (particle ranges per thread, per-thread rho
copies summed in thread order): per-particle results are identical to the
sequential code, the deposit agrees to rounding with the exact total kept, and a
given thread count is deterministic (no GPU)."""

import numpy as np
import pytest

from workloads import plasma


@pytest.fixture
def threaded(orc):
    yield orc
    orc.set_threads(1)


@pytest.mark.parametrize("ndim,n", [(1, (257,)), (2, (64, 48)), (3, (12, 10, 9))])
def test_threaded_particle_loops_match_sequential(threaded, ndim, n):
    orc = threaded
    w = plasma.maxwellian_box(ndim, n, ppc=12, nv=3, seed=120 + ndim)
    ref = orc.Simulation(ndim, w.n, w.dx, w.dt, weight=w.weight, B0=(0.0, 0.3, 0.9),
                         rtol=1e-12).load(w.x, w.v)
    ref.step(2)
    for T in (3, 8):
        orc.set_threads(T)
        assert orc.get_threads() == T
        sim = orc.Simulation(ndim, w.n, w.dx, w.dt, weight=w.weight, B0=(0.0, 0.3, 0.9),
                             rtol=1e-12).load(w.x, w.v)
        sim.step(2)
        # rho differs from the sequential sum by rounding only; the rest follows it
        assert np.abs(sim.rho_e - ref.rho_e).max() <= 1e-12 * np.abs(ref.rho_e).max()
        assert abs(sim.rho_e.sum() - ref.rho_e.sum()) <= 1e-9 * np.abs(ref.rho_e).sum()
        assert np.abs(sim.x - ref.x).max() <= 1e-9
        assert np.abs(sim.v - ref.v).max() <= 1e-9
        orc.set_threads(1)
    # per-particle loops alone are bit-identical
    E = np.random.default_rng(5).standard_normal(ndim * w.cells)
    orc.set_threads(1)
    g1 = orc.gather(ndim, w.n, w.dx, w.x, E)
    orc.set_threads(8)
    g8 = orc.gather(ndim, w.n, w.dx, w.x, E)
    np.testing.assert_array_equal(g1, g8)
    # determinism for a given thread count
    r8a = orc.deposit(ndim, w.n, w.dx, w.x, -0.5)
    r8b = orc.deposit(ndim, w.n, w.dx, w.x, -0.5)
    np.testing.assert_array_equal(r8a, r8b)
