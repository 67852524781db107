"""The 3D electromagnetic step (Sec. 2.2 E_Maxwell: 3D Yee FDTD with the Esirkepov
current and trilinear staggered gathers) on the GPU against the FP64 oracle's
EmSimulation3: particle state, E, B and rho within 1e-5 over ten steps with sorts,
Gauss's law and div B = 0 on the GPU fields, exact charge."""

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
    sim = oracle.EmSimulation3(n, dx, dt, c=c, weight=w.weight, B0=B0).load(w.x, w.v)
    ident = g.get_perm().copy()
    for k in range(1, 11):
        g.step(1)
        sim.step(1)
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    _, _, v, x = g.get_particles()
    L = np.asarray(w.L[:3])
    dist = np.abs(x - sim.x[ident])
    dist = np.minimum(dist, L - dist) / np.asarray(dx)
    assert dist.max() <= TOL, dist.max()
    assert rel(v, sim.v[ident], np.abs(sim.v).max()) <= TOL
    E, B = g.get_E(), g.get_B()
    assert rel(E, sim.E.ravel(), np.abs(sim.E).max()) <= TOL
    assert rel(B, sim.B.ravel(), np.abs(sim.B).max()) <= TOL
    rho = g.get_rho()
    rho_e = oracle.deposit(3, n, dx, sim.x, -1.0 * w.weight)
    assert rel(rho, sim.rho, np.abs(rho_e).max()) <= TOL
    # Gauss's law and div B = 0 on the GPU fields, to the FP32 rounding of the fields
    div = oracle.yee3_div_e(n, dx, E.reshape(3, -1))
    assert np.abs(div - rho).max() <= 1e-4 * np.abs(rho).max()
    divb = oracle.yee3_div_b(n, dx, B.reshape(3, -1))
    assert np.abs(divb).max() <= 1e-4 * max(np.abs(B).max(), 1e-30) / min(dx)
    d = g.get_diag()
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    assert d["error_flags"] == 0
    mw = w.m * w.weight
    scale = mw * np.abs(sim.v).sum()
    assert np.abs(np.asarray(d["momentum"]) - oracle.momentum(sim.v, mw)).max() <= TOL * scale
    g.close()
