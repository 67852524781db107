"""The Higuera-Cary pusher in the fused particle pass against the FP64 oracle's
(Sec. 2.2 A_Pusher lists it beside Boris): the same 1e-5 bars on momentum,
position, rho and E, and its distinguishing property, the exact relativistic
E x B drift, on the GPU."""

import math

import numpy as np
import pytest

import oracle
from workloads import plasma

pytestmark = pytest.mark.gpu
TOL = 1e-5
HC = 1


@pytest.fixture(scope="module")
def pk():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2608_15249_b300 as pk
    pk.lib()
    return pk


def _pair(pk, w, c, **over):
    """The workload's velocities are read as momenta per mass u (|u| ~ v_te, so the
    plasma is mildly relativistic for c of a few v_te)."""
    g = pk.from_workload(w, pusher=HC, c_light=c, cg_rtol=1e-7, **over)
    sim = oracle.Simulation(w.ndim, w.n, w.dx, w.dt, q=w.q, m=w.m, weight=w.weight, B0=w.B0,
                            E0=w.E0, rtol=1e-12, pusher="hc", c=c)
    return g, sim


def rel(a, b, d):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / d


@pytest.mark.parametrize("name,c", [("3d_mag", 3.0), ("2d3v_mag", 2.0), ("1d", 4.0)])
def test_hc_ten_steps_match_oracle(pk, name, c):
    w = {
        "3d_mag": plasma.magnetized_3d(n=(16, 12, 10), ppc=8, seed=61),
        "2d3v_mag": plasma.maxwellian_box(2, (32, 24), ppc=12, nv=3, dt=0.05, seed=62,
                                          B0=(0.0, 0.0, 2.0)),
        "1d": plasma.maxwellian_box(1, (97,), ppc=40, nv=1, dt=0.1, seed=63),
    }[name]
    g, sim = _pair(pk, w, c, sort_every=3)
    g.load(w.x, w.v)
    sim.load(w.x, w.v)
    ident = g.get_perm().copy()
    for k in range(1, 11):
        g.step(1)
        sim.step(1)
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    _, _, u, x = g.get_particles()
    L = np.asarray(w.L[: w.ndim])
    dist = np.abs(x - sim.x[ident])
    dist = np.minimum(dist, L - dist) / np.asarray(w.dx[: w.ndim])
    assert dist.max() <= TOL
    assert rel(u, sim.v[ident], np.abs(sim.v).max()) <= TOL
    assert rel(g.get_rho(), sim.rho, np.abs(sim.rho_e).max()) <= TOL
    assert rel(g.get_E(), sim.E, np.abs(sim.E).max()) <= TOL
    d = g.get_diag()
    assert abs(d["kinetic"] - sim.ke) <= 1e-5 * sim.ke
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    g.close()


def test_hc_relativistic_ExB_drift_on_gpu(pk):
    """Test particles (negligible weight) moving at the relativistic E x B drift in
    uniform crossed E0, B0 stay at it; with Boris they would gyrate."""
    c, Ey, Bz = 1.0, 0.5, 1.0
    vd = Ey / Bz
    ud = vd / math.sqrt(1.0 - vd * vd / c ** 2)
    n = 64
    x = np.column_stack([np.linspace(0.5, 15.5, n), np.linspace(0.3, 7.3, n),
                         np.linspace(0.1, 7.9, n)])
    u = np.tile([ud, 0.0, 0.0], (n, 1))
    cfg = pk.make_config(3, (16, 8, 8), dt=0.5, weight=1e-12, E0=(0.0, Ey, 0.0),
                         B0=(0.0, 0.0, Bz), nv=3, sort_every=0, pusher=HC, c_light=c)
    g = pk.Pic(cfg)
    g.load(x, u, half_push=False)
    g.step(20)
    _, _, un, _ = g.get_particles(positions=False)
    assert np.abs(un - u).max() <= 2e-6 * ud
    g.close()


def test_hc_nonrelativistic_limit_matches_boris(pk):
    """c = 0 (infinite) reduces the Higuera-Cary step to Boris up to FP32 rounding."""
    w = plasma.magnetized_3d(n=(16, 12, 10), ppc=8, seed=64)
    a = pk.from_workload(w, pusher=HC, c_light=0.0).load(w.x, w.v)
    b = pk.from_workload(w).load(w.x, w.v)
    a.step(3)
    b.step(3)
    ua, ub = a.get_particles(positions=False)[2], b.get_particles(positions=False)[2]
    assert np.abs(ua - ub).max() <= 1e-5 * np.abs(ub).max()
    a.close()
    b.close()
