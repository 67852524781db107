"""The 3D electromagnetic step (Sec. 2.2 E_Maxwell: 3D Yee FDTD with the Esirkepov
current and trilinear staggered gathers) on the GPU against the FP64 oracle's
EmSimulation3: particle state, E, B and rho within 1e-5 over ten steps with sorts,
Gauss's law and div B = 0 on the GPU fields, exact charge.  A dense cluster in a dilute
background sends particles through both paths of the particle step: the tiles' shared-
memory deposit windows and the global-memory kernel for the particles outside them."""

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


CASES = {
    "cubic": ((12, 10, 8), (1.0, 1.0, 1.0), 6, 3.0, (0.0, 0.0, 0.0), 0.1),
    "anisotropic_B0": ((10, 12, 9), (1.0, 0.8, 1.2), 8, 2.5, (0.2, -0.1, 0.7), 0.1),
    "many_blocks": ((24, 24, 24), (1.0, 1.0, 1.0), 40, 3.0, (0.0, 0.3, 0.5), 0.1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_em3_ten_steps_match_oracle(pk, name):
    n, dx, ppc, c, B0, dt = CASES[name]
    w = plasma.maxwellian_box(3, n, ppc=ppc, nv=3, dt=dt, seed=131, dx=dx)
    g = pk.from_workload(w, em=1, c_light=c, B0=B0, sort_every=3, cg_rtol=1e-7)
    g.load(w.x, w.v)
    _ten_steps_against_oracle(pk, g, n, dx, dt, c, B0, w.x, w.v, w.weight, w.m, w.np_)


# The particle kernel's deposit window, restated on the host: tiles of 256 consecutive
# (sorted) particles; a particle is in its tile's window when its old cell, relative
# to the old cell of the tile's middle particle (unwrapped to [-n/2, n/2]), lies in
# [1 - L, W - 3 - L] on every axis, W = (16, 16, 12) nodes, L = (7, 7, 5).
WIN, WIN_LO, TILE = np.array([16, 16, 12]), np.array([7, 7, 5]), 256


def window_split(cell, n):
    n = np.asarray(n)
    c = np.stack([cell % n[0], (cell // n[0]) % n[1], cell // (n[0] * n[1])], 1)
    inside = np.zeros(len(c), bool)
    for first in range(0, len(c), TILE):
        d = c[first:first + TILE] - c[min(first + TILE // 2, len(c) - 1)]
        d = np.where(2 * d > n, d - n, d)
        d = np.where(2 * d < -n, d + n, d)
        lc = d + WIN_LO
        inside[first:first + TILE] = ((lc >= 1) & (lc <= WIN - 3)).all(1)
    return inside


def test_em3_cluster_in_dilute_background_takes_both_paths(pk):
    """A Maxwellian cluster (20,000 electrons, Gaussian of 1.5 cells) in a uniform dilute
    background (0.25 per cell) on 40 x 36 x 28 cells, weight 2e-3: at load, the cluster's tiles lie
    in their windows and most background particles do not (checked with the host
    restatement of the window rule on the GPU's sorted state); ten steps with sorts
    match the oracle as in the uniform cases."""
    n, dx, c, B0, dt = (40, 36, 28), (1.0, 1.0, 1.0), 3.0, (0.0, 0.2, 0.4), 0.1
    rng = np.random.default_rng(77)
    L = np.asarray(n, float)
    bg = rng.uniform(0.0, 1.0, (int(0.25 * np.prod(n)), 3)) * L
    cl = (rng.normal(0.0, 1.5, (20000, 3)) + L / 2) % L
    x = np.concatenate([bg, cl])
    v = rng.normal(0.0, 1.0, x.shape)
    # a small weight keeps the cluster's own field weak (moves stay under a cell a step)
    weight = 2e-3
    cfg = pk.make_config(3, n, dx=dx, dt=dt, weight=weight, nv=3, B0=B0, em=1, c_light=c,
                         sort_every=3, cg_rtol=1e-7)
    g = pk.Pic(cfg).load(x, v)
    cell = g.get_particles(positions=False)[0]
    inside = window_split(cell, n)
    assert inside.sum() > 10000 and (~inside).sum() > 1000, (inside.sum(), (~inside).sum())
    _ten_steps_against_oracle(pk, g, n, dx, dt, c, B0, x, v, weight, 1.0, len(x))


def _ten_steps_against_oracle(pk, g, n, dx, dt, c, B0, x0, v0, weight, m, np_):
    sim = oracle.EmSimulation3(n, dx, dt, c=c, weight=weight, B0=B0).load(x0, v0)
    ident = g.get_perm().copy()
    for k in range(1, 11):
        g.step(1)
        sim.step(1)
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    _, _, v, x = g.get_particles()
    L = np.asarray(n, float) * np.asarray(dx)
    dist = np.abs(x - sim.x[ident])
    dist = np.minimum(dist, L - dist) / np.asarray(dx)
    assert dist.max() <= TOL, dist.max()
    assert rel(v, sim.v[ident], np.abs(sim.v).max()) <= TOL
    E, B = g.get_E(), g.get_B()
    assert rel(E, sim.E.ravel(), np.abs(sim.E).max()) <= TOL
    assert rel(B, sim.B.ravel(), np.abs(sim.B).max()) <= TOL
    rho = g.get_rho()
    rho_e = oracle.deposit(3, n, dx, sim.x, -1.0 * weight)
    assert rel(rho, sim.rho, np.abs(rho_e).max()) <= TOL
    # Gauss's law and div B = 0 on the GPU fields, to the FP32 rounding of the fields
    div = oracle.yee3_div_e(n, dx, E.reshape(3, -1))
    assert np.abs(div - rho).max() <= 1e-4 * np.abs(rho).max()
    divb = oracle.yee3_div_b(n, dx, B.reshape(3, -1))
    assert np.abs(divb).max() <= 1e-4 * max(np.abs(B).max(), 1e-30) / min(dx)
    d = g.get_diag()
    assert d["charge_fx_sum"] == np_ * (1 << d["fx_bits"])
    assert d["error_flags"] == 0
    mw = m * weight
    scale = mw * np.abs(sim.v).sum()
    assert np.abs(np.asarray(d["momentum"]) - oracle.momentum(sim.v, mw)).max() <= TOL * scale
    g.close()
