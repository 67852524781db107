"""The electromagnetic step (Sec. 2.2 E_Maxwell: Yee FDTD, with the Esirkepov current
and the staggered gathers) on the GPU against the FP64 oracle's EmSimulation: particle
state, E, B and rho within 1e-5 over ten steps with sorts, and Gauss's law kept."""

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


def rel(a, b, d):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / d


@pytest.mark.parametrize("n,dx,c,B0", [((32, 24), (1.0, 1.0), 3.0, (0.0, 0.0, 0.0)),
                                       ((40, 18), (0.5, 0.75), 2.0, (0.2, -0.1, 0.6))])
def test_em_ten_steps_match_oracle(pk, n, dx, c, B0):
    dt = 0.1
    w = plasma.maxwellian_box(2, n, ppc=10, nv=3, dt=dt, seed=81, dx=dx)
    g = pk.from_workload(w, em=1, c_light=c, B0=B0, sort_every=3, cg_rtol=1e-7)
    g.load(w.x, w.v)
    sim = oracle.EmSimulation(n, dx, dt, c=c, weight=w.weight, B0=B0).load(w.x, w.v)
    ident = g.get_perm().copy()
    for k in range(1, 11):
        g.step(1)
        sim.step(1)
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    _, _, v, x = g.get_particles()
    L = np.asarray(w.L[:2])
    dist = np.abs(x - sim.x[ident])
    dist = np.minimum(dist, L - dist) / np.asarray(dx)
    assert dist.max() <= TOL
    assert rel(v, sim.v[ident], np.abs(sim.v).max()) <= TOL
    E, B = g.get_E(), g.get_B()
    assert rel(E, sim.E.ravel(), np.abs(sim.E).max()) <= TOL
    assert rel(B, sim.B.ravel(), np.abs(sim.B).max()) <= TOL
    rho = g.get_rho()
    rho_e = oracle.deposit(2, n, dx, sim.x, -1.0 * w.weight)
    assert rel(rho, sim.rho, np.abs(rho_e).max()) <= TOL
    # Gauss's law on the GPU field: div E = rho up to the FP32 rounding of E
    div = oracle.yee_div_e(n, dx, E.reshape(3, -1))
    assert np.abs(div - rho).max() <= 1e-4 * np.abs(rho).max()
    d = g.get_diag()
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    g.close()


def test_em_rejects_unsupported_configurations(pk):
    w = plasma.maxwellian_box(2, (16, 16), ppc=2, nv=3, dt=0.1, seed=82)
    for bad in (dict(em=1, c_light=0.0), dict(em=1, c_light=20.0), dict(em=1, c_light=2.0, nv=2)):
        with pytest.raises(pk.PicError):
            pk.from_workload(w, **bad)


def _window_fits(cells, n, tile=256, cap=1024):
    """Per tile of the (sorted) particle order: does the tile's window (the box of its
    old cells relative to its first particle's cell, widened by one node below and
    two above) fit the kernel's shared-memory capacity?  The rule of the tiled
    kernel, restated here to check that a test case exercises both of its paths."""
    out = []
    for s in range(0, len(cells), tile):
        c = cells[s:s + tile]
        cx, cy = c % n[0], c // n[0]
        d = []
        for a, ca in ((0, cx), (1, cy)):
            dd = ca - ca[0]
            dd = np.where(2 * dd > n[a], dd - n[a], dd)
            dd = np.where(2 * dd < -n[a], dd + n[a], dd)
            d.append(dd)
        w0 = d[0].max() - d[0].min() + 4
        w1 = d[1].max() - d[1].min() + 4
        out.append(w0 <= cap and w1 <= cap and w0 * w1 <= cap)
    return np.array(out)


def test_em_windowed_and_spread_tiles_match_oracle(pk):
    """A dense cluster (tiles whose stencils fit the shared-memory windows) in a
    dilute background (tiles too spread out, taken particle by particle): both paths
    against the oracle over five steps, without re-sorting."""
    n, dx, c, dt = (64, 48), (1.0, 1.0), 3.0, 0.1
    rng = np.random.default_rng(83)
    L = np.array([n[0] * dx[0], n[1] * dx[1]])
    bg = rng.uniform(0.0, 1.0, (1500, 2)) * L
    cl = np.array([20.0, 30.0]) + rng.uniform(0.0, 4.0, (3000, 2))
    x = np.concatenate([bg, cl])
    v = rng.normal(0.0, 1.0, (x.shape[0], 3))
    weight = 0.02  # a light plasma: the cluster's own field stays well below a cell per step
    cfg = pk.make_config(2, n, dx=dx, dt=dt, nv=3, weight=weight, em=1, c_light=c,
                         sort_every=0, cg_rtol=1e-7)
    g = pk.Pic(cfg).load(x, v)
    sim = oracle.EmSimulation(n, dx, dt, c=c, weight=weight).load(x, v)
    perm = g.get_perm().copy()
    cell, _, _, _ = g.get_particles(positions=False)
    fits = _window_fits(np.asarray(cell, np.int64), n)
    assert fits.any() and not fits.all(), fits
    for _ in range(5):
        v_prev = sim.v.copy()
        g.step(1)
        sim.step(1)
    _, _, vg, xg = g.get_particles()
    dist = np.abs(xg - sim.x[perm])
    dist = np.minimum(dist, L - dist) / np.asarray(dx)
    assert dist.max() <= TOL
    assert rel(vg, sim.v[perm], np.abs(sim.v).max()) <= TOL
    assert rel(g.get_E(), sim.E.ravel(), np.abs(sim.E).max()) <= TOL
    assert rel(g.get_B(), sim.B.ravel(), np.abs(sim.B).max()) <= TOL
    rho_e = oracle.deposit(2, n, dx, sim.x, -1.0 * weight)
    assert rel(g.get_rho(), sim.rho, np.abs(rho_e).max()) <= TOL
    d = g.get_diag()
    assert d["charge_fx_sum"] == x.shape[0] * (1 << d["fx_bits"])
    # kinetic energy time-centred at the last push, summed over both kernels' slots
    ke_o = 0.5 * (0.5 * weight * float(np.sum(v_prev ** 2)) + 0.5 * weight * float(np.sum(sim.v ** 2)))
    assert abs(d["kinetic"] - ke_o) <= 1e-5 * ke_o
    g.close()
