"""Null-collision Monte Carlo (Sec. 2.2 G_collision) on the GPU against the FP64
oracle: the same counter-based draws keyed by particle id, so the same particles
collide with the same processes and angles; momenta and positions within 1e-5,
collision counts equal, charge exact, through sorts that move the particles."""

import numpy as np
import pytest

import oracle
from workloads import plasma

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def pk():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2608_15249_b300 as pk
    pk.lib()
    return pk


P = dict(density=1.0, sigma_el=0.4, sigma_exc=0.15, eps_exc=0.8, mass_ratio=1e-3, vmax=5.0,
         seed=2024)


def rel(a, b, d):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / d


def _pair(pk, w, **over):
    g = pk.from_workload(w, cg_rtol=1e-7, **over)
    g.set_collisions(**P)
    sim = oracle.Simulation(w.ndim, w.n, w.dx, w.dt, q=w.q, m=w.m, weight=w.weight, B0=w.B0,
                            E0=w.E0, rtol=1e-12, collisions=P)
    return g, sim


@pytest.mark.parametrize("name", ["1d3v", "2d3v", "3d"])
def test_mcc_ten_steps_match_oracle(pk, name):
    w = {
        "1d3v": plasma.maxwellian_box(1, (97,), ppc=60, nv=3, dt=0.1, seed=71),
        "2d3v": plasma.maxwellian_box(2, (40, 36), ppc=16, nv=3, dt=0.1, seed=72),
        "3d": plasma.maxwellian_box(3, (16, 12, 10), ppc=8, nv=3, dt=0.1, seed=73),
    }[name]
    g, sim = _pair(pk, w, sort_every=3)
    g.load(w.x, w.v)
    sim.load(w.x, w.v)
    ident = g.get_perm().copy()
    total = np.zeros(3, np.int64)
    for k in range(1, 11):
        g.step(1)
        sim.step(1)
        d = g.get_diag()
        np.testing.assert_array_equal(d["mcc_counts"], sim.mcc_counts)
        total += sim.mcc_counts
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    assert total[0] > 50 and total[1] > 5
    _, _, v, x = g.get_particles()
    L = np.asarray(w.L[: w.ndim])
    dist = np.abs(x - sim.x[ident])
    dist = np.minimum(dist, L - dist) / np.asarray(w.dx[: w.ndim])
    assert dist.max() <= TOL
    assert rel(v, sim.v[ident], np.abs(sim.v).max()) <= TOL
    assert rel(g.get_rho(), sim.rho, np.abs(sim.rho_e).max()) <= TOL
    assert rel(g.get_E(), sim.E, np.abs(sim.E).max()) <= TOL
    d = g.get_diag()
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    g.close()


def test_collide_alone_matches_oracle(pk):
    """One collision pass on the loaded (sorted) state, against the oracle's on the
    same particles in load order."""
    w = plasma.maxwellian_box(2, (32, 24), ppc=20, nv=3, dt=0.1, seed=74)
    g, sim = _pair(pk, w)
    g.load(w.x, w.v, half_push=False)
    sim.load(w.x, w.v, half_push=False)
    g.collide()
    counts = sim.collide()
    np.testing.assert_array_equal(g.get_diag()["mcc_counts"], counts)
    perm = g.get_perm()
    _, _, v, _ = g.get_particles(positions=False)
    assert rel(v, sim.v[perm], np.abs(sim.v).max()) <= TOL
    g.close()


def test_collisions_are_deterministic_and_off_by_default(pk):
    w = plasma.maxwellian_box(1, (64,), ppc=30, nv=3, dt=0.1, seed=75)
    runs = []
    for _ in range(2):
        g = pk.from_workload(w).set_collisions(**P).load(w.x, w.v)
        g.step(4)
        runs.append(g.get_particles(positions=False)[2])
        g.close()
    np.testing.assert_array_equal(runs[0], runs[1])
    g = pk.from_workload(w).load(w.x, w.v)
    g.step(1)
    assert g.get_diag()["mcc_counts"] == [0, 0, 0]
    with pytest.raises(pk.PicError):
        g.collide()
    g.close()
