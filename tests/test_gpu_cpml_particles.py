"""Particles in the non-periodic electromagnetic mode (Sec. 2.2 E_Maxwell with the
convolutional PML; conducting walls, absorbing particle walls) on the GPU against
the FP64 oracle's CpmlPlasma: particle state, E, B and the electron charge within
1e-5 while particles reach the layer and are absorbed, the same particles absorbed,
the interior Gauss invariant kept on the GPU fields, and positions outside the box
rejected at load."""

import numpy as np
import pytest

import oracle

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


def _gpu(pk, n, dx, dt, c, npml, weight, B0, npart):
    cfg = pk.make_config(2, n, dx=dx, dt=dt, weight=weight, B0=B0, nv=3, em=1, c_light=c,
                         em_boundary=1, pml_cells=npml, sort_every=1, rho_background=0.0)
    return pk.Pic(cfg)


def _interior(n, margin):
    j, i = np.meshgrid(np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return ((i >= margin) & (i < n[0] - margin) & (j >= margin) & (j < n[1] - margin)).ravel()


def _div_e(n, dx, E):
    ex = E[0].reshape(n[1], n[0])
    ey = E[1].reshape(n[1], n[0])
    ddx = ex - np.pad(ex, ((0, 0), (1, 0)))[:, :-1]
    ddy = ey - np.pad(ey, ((1, 0), (0, 0)))[:-1, :]
    return (ddx / dx[0] + ddy / dx[1]).ravel()


def test_plasma_with_absorbing_walls_matches_oracle(pk):
    rng = np.random.default_rng(11)
    n, dx, dt, c, npml = (40, 36), (1.0, 0.9), 0.1, 2.0, 6
    box = np.array([(n[0] - 1) * dx[0], (n[1] - 1) * dx[1]])
    x = 2.0 + rng.uniform(0, 1, (3000, 2)) * (box - 4.0)
    v = rng.normal(0, 1.5, (3000, 3))
    B0 = (0.0, 0.0, 0.4)
    g = _gpu(pk, n, dx, dt, c, npml, 0.05, B0, len(x))
    g.load(x, v)
    sim = oracle.CpmlPlasma(n, dx, dt, c, npml, weight=0.05, B0=B0).load(x, v)
    ident = g.get_perm().copy()
    inner = _interior(n, npml + 2)
    E0 = g.get_E().reshape(3, -1)
    d0 = _div_e(n, dx, E0) - g.get_rho()
    for _ in range(40):
        g.step(1)
        sim.step(1)
        ident = ident[g.get_perm()]  # a sort every step drops the absorbed
        assert len(ident) == sim.x.shape[0] == g.np
    assert sim.absorbed > 100
    # the same particles are left, in the same state
    row = np.full(len(x), -1)
    row[sim.ids] = np.arange(len(sim.ids))
    assert np.all(row[ident] >= 0)
    _, _, vg, xg = g.get_particles()
    xo, vo = sim.x[row[ident]], sim.v[row[ident]]
    assert np.abs(xg - xo).max() / min(dx) <= TOL
    assert rel(vg, vo, np.abs(vo).max()) <= TOL
    E, B = g.get_E().reshape(3, -1), g.get_B().reshape(3, -1)
    assert rel(E, sim.E, np.abs(sim.E).max()) <= TOL
    assert rel(B, sim.B, np.abs(sim.B).max()) <= TOL
    rho = g.get_rho()
    assert rel(rho, sim.rho, np.abs(sim.rho).max()) <= TOL
    # charge conservation away from the layer and the walls, on the GPU fields
    d1 = _div_e(n, dx, E) - rho
    assert np.abs(d1[inner] - d0[inner]).max() <= 1e-4 * np.abs(d0[inner]).max()
    d = g.get_diag()
    assert d["np"] == sim.x.shape[0] and d["error_flags"] == 0
    assert d["charge_fx_sum"] == d["np"] * (1 << d["fx_bits"])
    g.close()


def test_ballistic_particles_are_absorbed_when_they_leave(pk):
    """Test particles (negligible weight: no field of their own) move in straight lines
    and are dropped at the end of the step in which they leave the box, exactly as in
    the oracle's weightless run."""
    rng = np.random.default_rng(13)
    n, dx, dt, c, npml = (20, 16), (1.0, 1.0), 0.25, 1.0, 4
    box = np.array([19.0, 15.0])
    x = rng.uniform(0.5, 1.0, (400, 2)) * box
    v = rng.normal(0, 3.0, (400, 3))
    v[:, :2] = np.clip(v[:, :2], -3.8, 3.8)  # under one cell per step
    g = _gpu(pk, n, dx, dt, c, npml, 1e-12, (0.0, 0.0, 0.0), len(x))
    g.load(x, v, half_push=False)
    sim = oracle.CpmlPlasma(n, dx, dt, c, npml, weight=0.0).load(x, v, half_push=False)
    for _ in range(8):
        g.step(1)
        sim.step(1)
        assert g.np == sim.x.shape[0]
    assert sim.absorbed > 0
    g.close()


def test_load_outside_the_box_is_rejected(pk):
    n, dx = (20, 16), (1.0, 1.0)
    x = np.array([[5.0, 5.0], [19.2, 3.0]])  # the second past (n0 - 1) dx = 19
    v = np.zeros((2, 3))
    g = _gpu(pk, n, dx, 0.1, 1.0, 4, 0.1, (0.0, 0.0, 0.0), 2)
    with pytest.raises(pk.PicError) as ei:
        g.load(x, v)
    assert ei.value.status == -6
    g.close()
