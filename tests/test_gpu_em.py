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
