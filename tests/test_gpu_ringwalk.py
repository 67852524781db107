"""Parity with the FP64 oracle at sizes where every persistent CTA of the particle
kernels walks its tile ring several times (more tiles than resident CTAs x ring
stages): stage reuse, the barrier parity flip, the charge-window reset between
tiles and the wait for a stage's bulk store before its refill all run.  The
smaller parity cases elsewhere give each CTA at most one tile.

Each case runs ten cycles with sorts and checks, besides positions, velocities,
rho and E (1e-5, the same denominators as the other parity tests), the total
momentum diagnostic m w sum v of the last push against the oracle's, on the scale
sum |m w v| (a Maxwellian's net momentum is itself near zero)."""

import dataclasses

import numpy as np
import pytest

import oracle
from workloads import plasma

pytestmark = pytest.mark.gpu
TOL = 1e-5
SMS = 148


@pytest.fixture(scope="module")
def pk():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2608_15249_b300 as pk
    pk.lib()
    return pk


def rel(a, b, d):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / d


def _walks_ring(np_, tile, ctas_per_sm, stages=3):
    """At least stages + 1 tiles for every resident CTA."""
    return np_ // tile >= (stages + 1) * SMS * ctas_per_sm


def _check_state(w, g, sim, ident, v_o=None, ill_conditioned=0):
    """Positions (wrapped, in cells) and velocities within TOL of the oracle's; with
    ill_conditioned > 0, up to that many particles may exceed TOL (but not 1e-3)."""
    _, _, v, x = g.get_particles()
    L = np.asarray(w.L[: w.ndim])
    dist = np.abs(x - sim.x[ident])
    dist = np.minimum(dist, L - dist) / np.asarray(w.dx[: w.ndim])
    vo = sim.v[ident] if v_o is None else v_o[ident]
    dv = np.abs(v - vo) / np.abs(vo).max()
    off = (dist.max(axis=1) > TOL) | (dv.max(axis=1) > TOL)
    assert off.sum() <= ill_conditioned, (off.sum(), dist.max(), dv.max())
    assert dist.max() <= (1e-3 if ill_conditioned else TOL), dist.max()
    assert dv.max() <= (1e-3 if ill_conditioned else TOL), dv.max()
    return int(off.sum())


def _check_momentum(d, P_oracle, v_o, mw):
    scale = mw * np.abs(v_o).sum()
    nv = v_o.shape[1]
    dP = np.abs(np.asarray(d["momentum"][:nv]) - np.asarray(P_oracle[:nv]))
    assert dP.max() <= TOL * scale, (d["momentum"], P_oracle, scale)


CASES = {
    # (workload, tile of the pass, resident CTAs per SM of the pass)
    "3d_mag_48": (lambda: plasma.magnetized_3d(n=(48, 48, 48), ppc=10, seed=91), 512, 3),
    "2d_512x320": (lambda: plasma.maxwellian_box(2, (512, 320), ppc=16, nv=2, seed=92), 512, 4),
    # (a 1D box of 1,024 cells: the FP32 potential's rounding, amplified by the
    # box length over the node spacing, stays below the 1e-5 bar on E)
    "1d3v_1024_E0": (lambda: dataclasses.replace(
        plasma.maxwellian_box(1, (1024,), ppc=2400, nv=3, seed=93), E0=(0.02, 0.0, 0.01)),
        512, 4),
}


@pytest.mark.parametrize("name", list(CASES))
def test_ring_walk_ten_steps(pk, name):
    make, tile, per_sm = CASES[name]
    w = make()
    assert _walks_ring(w.np_, tile, per_sm), w.np_
    g = pk.from_workload(w, sort_every=3, cg_rtol=1e-7, solver=pk.AP_PIC_SOLVER_FFT)
    g.load(w.x, w.v)
    sim = oracle.Simulation(w.ndim, w.n, w.dx, w.dt, q=w.q, m=w.m, weight=w.weight, B0=w.B0,
                            E0=w.E0, rtol=1e-12).load(w.x, w.v)
    ident = g.get_perm().copy()
    for k in range(1, 11):
        g.step(1)
        sim.step(1)
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    _check_state(w, g, sim, ident)
    assert rel(g.get_rho(), sim.rho, np.abs(sim.rho_e).max()) <= TOL
    assert rel(g.get_E(), sim.E, np.abs(sim.E).max()) <= TOL
    d = g.get_diag()
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    assert d["error_flags"] == 0
    assert abs(d["kinetic"] - sim.ke) <= TOL * sim.ke
    _check_momentum(d, sim.momentum(), sim.v, w.m * w.weight)
    g.close()


def test_ring_walk_higuera_cary(pk):
    """The relativistic pusher's mode of the pass (c = 3 v_te, B0 = 2 z) at 2.36M
    particles; its momentum diagnostic sums u = gamma v."""
    w = plasma.maxwellian_box(2, (256, 256), ppc=36, nv=3, dt=0.05, B0=(0.0, 0.0, 2.0),
                              seed=94)
    assert _walks_ring(w.np_, 512, 4)
    c = 3.0
    g = pk.from_workload(w, pusher=pk.AP_PIC_PUSHER_HIGUERA_CARY, c_light=c, sort_every=3,
                         solver=pk.AP_PIC_SOLVER_FFT).load(w.x, w.v)
    sim = oracle.Simulation(2, w.n, w.dx, w.dt, weight=w.weight, B0=w.B0, rtol=1e-12,
                            pusher="hc", c=c).load(w.x, w.v)
    ident = g.get_perm().copy()
    for k in range(1, 11):
        g.step(1)
        sim.step(1)
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    _check_state(w, g, sim, ident)
    assert rel(g.get_E(), sim.E, np.abs(sim.E).max()) <= TOL
    d = g.get_diag()
    assert abs(d["kinetic"] - sim.ke) <= TOL * sim.ke
    _check_momentum(d, sim.momentum(), sim.v, w.weight)
    g.close()


def test_ring_walk_collisions(pk):
    """The null-collision pass after the particle pass on 2.36M electrons: equal
    collision counts every step; the diagnostic momentum is that of the push, taken
    before the collisions of the step.

    An excitation just above its threshold leaves the speed sqrt(v^2 - 2 eps / m):
    there the FP32 state's rounding of v^2 (relative 1e-7, present before the
    collision) is amplified by v^2 / (2 delta), delta = v^2 - 2 eps / m.  Over the
    ~1M collisions of this run a few such particles end up a few 1e-5 away from the
    oracle; at most 1e-5 N particles may exceed the bar, none by more than 1e-3."""
    P = dict(density=1.0, sigma_el=0.3, sigma_exc=0.1, eps_exc=0.8, mass_ratio=1e-3, vmax=6.0,
             seed=77)
    w = plasma.maxwellian_box(2, (256, 256), ppc=36, nv=3, dt=0.1, seed=95)
    g = pk.from_workload(w, sort_every=3, solver=pk.AP_PIC_SOLVER_FFT)
    g.set_collisions(**P)
    g.load(w.x, w.v)
    sim = oracle.Simulation(2, w.n, w.dx, w.dt, weight=w.weight, rtol=1e-12,
                            collisions=P).load(w.x, w.v)
    ident = g.get_perm().copy()
    mw = w.m * w.weight
    for k in range(1, 11):
        g.step(1)
        # the oracle's step, split so that the momentum of the push can be read
        sim.push()
        v_push = sim.v.copy()
        sim.move()
        sim.collide()
        sim.update_field()
        sim.t += sim.dt
        sim.step_count += 1
        d = g.get_diag()
        np.testing.assert_array_equal(d["mcc_counts"], sim.mcc_counts)
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    assert int(np.sum(sim.mcc_counts)) > 0
    _check_state(w, g, sim, ident, ill_conditioned=max(1, int(1e-5 * w.np_)))
    _check_momentum(d, oracle.momentum(v_push, mw), v_push, mw)
    g.close()


def test_ring_walk_electromagnetic(pk):
    """The electromagnetic particle kernels (256-particle tiles) on 786k electrons of a
    2D3V Maxwellian with B0: state, E, B within 1e-5 of the oracle's EmSimulation
    after ten steps with sorts, and the momentum of the last push."""
    n, dx, c, B0 = (128, 128), (1.0, 1.0), 3.0, (0.1, 0.0, 0.5)
    w = plasma.maxwellian_box(2, n, ppc=48, nv=3, dt=0.1, seed=96)
    assert _walks_ring(w.np_, 256, 4, stages=4)
    g = pk.from_workload(w, em=1, c_light=c, B0=B0, sort_every=3, cg_rtol=1e-7)
    g.load(w.x, w.v)
    sim = oracle.EmSimulation(n, dx, w.dt, c=c, weight=w.weight, B0=B0).load(w.x, w.v)
    ident = g.get_perm().copy()
    for k in range(1, 11):
        g.step(1)
        sim.step(1)
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    _check_state(w, g, sim, ident)
    assert rel(g.get_E(), sim.E.ravel(), np.abs(sim.E).max()) <= TOL
    assert rel(g.get_B(), sim.B.ravel(), np.abs(sim.B).max()) <= TOL
    d = g.get_diag()
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    _check_momentum(d, oracle.momentum(sim.v, w.m * w.weight), sim.v, w.m * w.weight)
    g.close()
