"""Parity at the benchmark's full size and launch configuration (2D two-stream,
512 x 512 nodes, 64 electrons per cell, 16,777,216 electrons, the persistent particle
pass as bench.py launches it): rho and E on the whole grid, the exact charge, the
bit-exact cells and sort permutation at load, and one full step of a random sample of
particles against the oracle's; plus empty loads."""

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def pk():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2608_15249_b300 as pk
    pk.lib()
    return pk


def test_full_size_two_stream_against_oracle(pk):
    w = workloads.two_stream_2d(n=(512, 512), ppc=64, seed=2)
    g = pk.from_workload(w, cg_rtol=1e-7)
    g.load(w.x, w.v)
    sim = oracle.Simulation(2, w.n, w.dx, w.dt, weight=w.weight, rtol=1e-10).load(w.x, w.v)
    d = g.get_diag()
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    rho_e = np.abs(sim.rho_e).max()
    assert np.abs(g.get_rho() - sim.rho).max() <= TOL * rho_e
    assert np.abs(g.get_E() - sim.E).max() <= TOL * np.abs(sim.E).max()
    # the load sorted: cells and permutation bit-exact
    perm = g.get_perm()
    cell_o, _ = sim.cells_offsets()
    brick = [g.cfg.brick[a] for a in range(2)]
    key = oracle.sort_key(2, w.n, brick, cell_o)
    np.testing.assert_array_equal(perm, oracle.counting_sort(key, oracle.num_keys(2, w.n, brick)))
    cell, _, _, _ = g.get_particles(positions=False)
    np.testing.assert_array_equal(cell, cell_o[perm])
    # one full step; a random sample of particles against the oracle's
    g.step(1)
    sim.step(1)
    rng = np.random.default_rng(0)
    sample = rng.choice(w.np_, 4096, replace=False)
    _, _, v, x = g.get_particles()
    xo, vo = sim.x[perm[sample]], sim.v[perm[sample]]
    L = np.asarray(w.L[:2])
    dist = np.abs(x[sample] - xo)
    dist = np.minimum(dist, L - dist)
    assert dist.max() <= TOL
    assert np.abs(v[sample] - vo).max() <= TOL * np.abs(sim.v).max()
    assert np.abs(g.get_rho() - sim.rho).max() <= TOL * rho_e
    assert np.abs(g.get_E() - sim.E).max() <= TOL * np.abs(sim.E).max()
    g.close()


@pytest.mark.parametrize("solver", [0, 1])
def test_empty_load_and_steps(pk, solver):
    """No particles: the load and steps run, the field stays zero, the charge is zero."""
    cfg = pk.make_config(2, (32, 24), dt=0.1, nv=2, solver=solver)
    g = pk.Pic(cfg).load(np.zeros((0, 2)), np.zeros((0, 2)))
    g.step(3)
    g.sort()
    d = g.get_diag()
    assert d["np"] == 0 and d["charge_fx_sum"] == 0 and d["step"] == 3
    assert np.abs(g.get_E()).max() == 0.0
    g.close()
